"""The surrogate's tensor-core GEMM (tcgen05, accumulator in tensor memory) against an FP64
product of the same bfloat16 operands, over the operand layouts the network uses (row-major
activations times [out][in] weights, and the transposed forms of the backward pass) and
sizes with ragged tails in M, N and K."""
import ctypes as C

import numpy as np
import pytest

from oracle import mlp as omlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bf16(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.cuda(), omlp.to_bf16(a)


@pytest.mark.parametrize("M,N,K,layout", [(128, 128, 64, "nt"), (200, 130, 100, "nt"),
                                          (4096, 256, 48, "nt"), (300, 48, 256, "nt"),
                                          (256, 48, 1000, "tn"), (513, 256, 48, "nn"),
                                          (7, 5, 3, "nt"), (128, 128, 0, "nt")])
def test_gemm_matches_fp64(M, N, K, layout):
    from paper_2605_18566_gb300 import _lib
    lib = _lib.load()
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    if layout == "nt":          # A [M][K] row-major, B given as [N][K] (weights [out][in])
        a = rng.normal(size=(M, K)); bt = rng.normal(size=(N, K))
        At, Ar = _bf16(a); Bt, Br = _bf16(bt)
        sam, sak, sbk, sbn = K, 1, 1, K
        ref = Ar @ Br.T
    elif layout == "tn":        # A given as [K][M] (dZ), B [K][N] (activations)
        at = rng.normal(size=(K, M)); b = rng.normal(size=(K, N))
        At, Ar = _bf16(at); Bt, Br = _bf16(b)
        sam, sak, sbk, sbn = 1, M, N, 1
        ref = Ar.T @ Br
    else:                       # A [M][K], B [K][N] row-major (dZ . W)
        a = rng.normal(size=(M, K)); b = rng.normal(size=(K, N))
        At, Ar = _bf16(a); Bt, Br = _bf16(b)
        sam, sak, sbk, sbn = K, 1, N, 1
        ref = Ar @ Br
    Cg = torch.full((M, N), float("nan"), device="cuda")
    flag = C.c_int(0)
    st = lib.hjg_gemm_bf16(C.c_void_p(At.data_ptr()), sam, sak, C.c_void_p(Bt.data_ptr()), sbk, sbn,
                           M, N, K, C.c_void_p(Cg.data_ptr()), N, C.byref(flag), None)
    assert st == 0 and flag.value == 0, (st, flag.value)
    got = Cg.cpu().numpy().astype(np.float64)
    tol = 1e-5 * np.sqrt(max(K, 1)) * (1 + np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol + 1e-6), np.abs(got - ref).max()
