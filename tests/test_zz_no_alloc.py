"""The allocation-free dose entry point (lgk_fetch_doses_device) against the
regular one (lgk_fetch_doses).

It serves callers that cannot allocate device memory at run time (memory owned
by another pool or arena, real-time loops, a GPU reserved up front): they pass
device buffers, and the call stages the plans' sector times in the library's
static device scratch instead of allocating.  This file is collected last so a
run that stops at the first failure has run every other test first; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

from oracle import lp as L
from oracle import metrics as M
from synth import cases as SC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk
    case = SC.workload_case(0)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(3)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    cs = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                         case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                         params=lgk.default_params(device=0))
    pts, _, _ = SC.eval_grid(case, spacing=2.0, margin=8.0)
    phi_eval = SC.dose_rate(pts, case.iso)
    return torch, lgk, cs, W, rho, phi_eval


def test_device_doses_match_fetch_doses_on_two_calls_in_a_row(env):
    torch, lgk, cs, W, rho, phi_eval = env
    phi_d = torch.from_numpy(phi_eval).to("cuda:0")
    # two calls in a row, different plans and batch sizes: the second must not
    # see anything of the first in the shared scratch
    for K, iters in ((9, 300), (4, 40)):
        res = lgk.solve_weightings(cs, W[:K], rho[:K], tol=0.0, max_iter=iters)
        ref = lgk.fetch_doses(res, phi_eval)
        out = torch.full((K, phi_eval.shape[0]), np.nan, dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        lgk.fetch_doses_device(res, phi_d.data_ptr(), phi_eval.shape[0], out.data_ptr())
        got = out.cpu().numpy()
        # same FP64 kernel on the same sector times: the tolerance of the
        # dose check in the parity tests
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        # and the oracle's dose d = Phi_eval t (FP64 on the host) from the
        # plans' sector times
        t, _ = lgk.fetch_times(res)
        np.testing.assert_allclose(got, M.dose(phi_eval, t.T).T, rtol=1e-12, atol=1e-12)


def test_device_doses_allocate_nothing(env):
    """The property the entry point exists for: after its first call on the
    device (which looks up the scratch array), a call leaves the device's
    free memory unchanged."""
    torch, lgk, cs, W, rho, phi_eval = env
    res = lgk.solve_weightings(cs, W[:3], rho[:3], tol=0.0, max_iter=20)
    phi_d = torch.from_numpy(phi_eval).to("cuda:0")
    out = torch.empty((3, phi_eval.shape[0]), dtype=torch.float64, device="cuda:0")
    torch.cuda.synchronize()
    lgk.fetch_doses_device(res, phi_d.data_ptr(), phi_eval.shape[0], out.data_ptr())
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(3):
        lgk.fetch_doses_device(res, phi_d.data_ptr(), phi_eval.shape[0], out.data_ptr())
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)


def test_device_doses_reject_host_buffers_and_oversized_batches(env):
    torch, lgk, cs, W, rho, phi_eval = env
    res = lgk.solve_weightings(cs, W[:2], rho[:2], tol=0.0, max_iter=5)
    out = torch.empty((2, phi_eval.shape[0]), dtype=torch.float64, device="cuda:0")
    with pytest.raises(lgk.LgkError) as e:          # a host pointer is refused, not used
        lgk.fetch_doses_device(res, phi_eval.ctypes.data, phi_eval.shape[0], out.data_ptr())
    assert e.value.code == 1
    # K x 24N beyond the static scratch is refused with a clear error: a small
    # case with 44 isocenters (24N = 1056) and K just past the limit
    small = SC.make_case([(np.zeros(3), np.full(3, 8.0))], n_target_pts=60, n_ring=20,
                         n_ld1=10, n_ld2=10, n_iso=44, seed=3)
    cs2 = lgk.create_case(small.phi, small.kind, small.struct_id, small.n_iso, small.d_presc,
                          small.q_area, small.q_vol, small.d_ld1, small.d_ld2, small.phi_cal,
                          params=lgk.default_params(device=0))
    K_big = lgk.LGK_NOALLOC_MAX_TIMES // (24 * small.n_iso) + 1
    assert K_big <= 4096
    Wb = np.tile(np.array([[1.0, 1.0, 0.5, 1e-3]]), (K_big, 1))
    big = lgk.solve_weightings(cs2, Wb, np.full(K_big, 100.0), tol=0.0, max_iter=1)
    phi_small = torch.from_numpy(np.ascontiguousarray(small.phi[:8])).to("cuda:0")
    dose_big = torch.empty((K_big, 8), dtype=torch.float64, device="cuda:0")
    with pytest.raises(lgk.LgkError) as e:
        lgk.fetch_doses_device(big, phi_small.data_ptr(), 8, dose_big.data_ptr())
    assert e.value.code == 1 and "scratch" in str(e.value)
