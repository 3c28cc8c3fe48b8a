"""GPU certificate (Cor. 2.9) against the oracle's definition.

The sweep writes each state's Monte-Carlo standard error sqrt(1/ESS - 1/N)/|c| with the
coefficient c that sweep used; the certificate kernel turns (v, se, ESS, the last sweep's
sup-norm change) into bands and labels.  Both are compared with the oracle's functions on
the GPU's own iterate (the iterate itself is covered by the parity tests), and the labels
of a full solve are compared with those of the oracle's FP64 trajectory."""
import numpy as np
import pytest

import hjg_inputs
import oracle
from helpers import problem_for, solver_for

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W1, W2 = hjg_inputs.DUBINS3, hjg_inputs.ROCKETS6


@pytest.mark.parametrize("w,M,N,K", [(W1, 4096, 4096, 4), (W2, 777, 16384, 3)], ids=["dubins3", "rockets6"])
def test_certificate_matches_oracle_definition(w, M, N, K):
    x = torch.from_numpy(hjg_inputs.points(w, M=M)).cuda()
    s = solver_for(w, N=N, K=K)
    s.set_points(x)
    s.picard_sweep(K - 1)
    c_used = s.get_state()["c"].cpu().numpy().astype(np.float64)
    r, sup = s.picard_sweep(1)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    e0, q, dp, ess_min = 0.01, 0.1, 0.05, 8.0
    lab, band, se, counts = s.certify(e0, q, dp, ess_min)
    lab, band, se = lab.cpu().numpy(), band.cpu().numpy(), se.cpu().numpy()
    s.close()
    se_ref = oracle.mc_std_error(st["ess"], c_used, N)
    # ESS is stored in FP32: bound the effect of its rounding on 1/ESS - 1/N
    var_tol = 2.0**-22 / st["ess"].astype(np.float64) / c_used**2
    assert np.all(np.abs(se.astype(np.float64)**2 - se_ref**2) <= 1e-5 * se_ref**2 + var_tol)
    lab_ref, band_ref = oracle.certify(st["v"], se, sup[-1], e0, q, dp, ess=st["ess"], ess_min=ess_min)
    np.testing.assert_allclose(band, band_ref, rtol=1e-6)
    tie = np.abs(np.abs(st["v"]) - band_ref) <= 1e-6 * (1.0 + band_ref)
    assert np.all((lab == lab_ref) | tie)
    assert counts == (int((lab == 1).sum()), int((lab == -1).sum()), int((lab == 0).sum()))
    assert counts[2] > 0 and counts[0] + counts[1] > 0


def test_certificate_labels_of_full_solve_vs_fp64_trajectory():
    """Labels from the GPU solve and from the oracle's own FP64 trajectory agree wherever
    the two values agree within the parity tolerance and are not within it of the band."""
    w, M, N, K = W1, 2048, 4096, 6
    xn = hjg_inputs.points(w, M=M)
    s = solver_for(w, N=N, K=K)
    s.set_points(torch.from_numpy(xn).cuda())
    r, sup = s.picard_sweep(K)
    st = {k: t.cpu().numpy() for k, t in s.get_state().items()}
    lab, band, se, counts = s.certify(0.0, 0.0, 0.05)
    lab, band = lab.cpu().numpy(), band.cpu().numpy()
    s.close()
    ref = oracle.picard(problem_for(w), xn.astype(np.float64), N, K)
    tol = 1e-4 * (1.0 + np.abs(ref["v"]))
    close = np.abs(st["v"] - ref["v"]) <= tol
    clear = np.abs(np.abs(ref["v"]) - band) > 2 * tol
    lab_ref = np.where(ref["v"] > band, 1, np.where(ref["v"] < -band, -1, 0))
    sel = close & clear
    assert sel.mean() > 0.9
    assert np.all(lab[sel] == lab_ref[sel])


def test_certify_needs_a_sweep():
    from paper_2605_18566_gb300 import HJGError
    s = solver_for(W1, N=256, K=1)
    s.set_points(torch.from_numpy(hjg_inputs.points(W1, M=64)).cuda())
    with pytest.raises(HJGError):
        s.certify()
    s.picard_sweep(1)
    s.certify()
    with pytest.raises(HJGError):
        s.certify(q=1.0)
    s.close()
