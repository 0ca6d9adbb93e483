"""GPU tests of the asynchronous solve (lgk_solve_weightings_async +
lgk_wait): the wait runs out on the host while the solve is still running
(no device wait is involved), results are refused until a wait succeeds, the
case is busy meanwhile, the results equal the blocking solve's bit for bit
(same arithmetic), and freeing a running result stops its solve."""
import time

import numpy as np
import pytest

from oracle import lp as L
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
                         case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal)
    return lgk, cs, W, rho


def test_async_solve_wait_times_out_then_matches_blocking_solve(env):
    lgk, cs, W, rho = env
    ref = lgk.fetch_stats(lgk.solve_weightings(cs, W, rho, tol=1e-4, max_iter=20000))
    res = lgk.solve_weightings_async(cs, W, rho, tol=1e-4, max_iter=20000)
    # the solve takes thousands of iterations: a 0 ms wait runs out on the host
    assert lgk.wait(res, 0) is False
    with pytest.raises(lgk.LgkError) as e:          # results refused until waited for
        lgk.fetch_stats(res)
    assert e.value.code == 1 and "lgk_wait" in str(e.value)
    with pytest.raises(lgk.LgkError) as e:          # the case is busy
        lgk.solve_weightings(cs, W, rho, tol=1e-4, max_iter=10)
    assert e.value.code == 1 and "busy" in str(e.value)
    assert lgk.wait(res, 600000) is True
    assert lgk.wait(res, 0) is True                 # waiting again is harmless
    got = lgk.fetch_stats(res)
    np.testing.assert_array_equal(got["iters"], ref["iters"])
    np.testing.assert_array_equal(got["obj"], ref["obj"])
    np.testing.assert_array_equal(got["converged"], ref["converged"])
    assert got["converged"].all()


def test_freeing_a_running_async_solve_stops_it(env):
    lgk, cs, W, rho = env
    res = lgk.solve_weightings_async(cs, W, rho, tol=0.0, max_iter=10 ** 6)
    assert lgk.wait(res, 50) is False
    t0 = time.time()
    res.close()                                     # cancels at the next graph replay
    assert time.time() - t0 < 30.0
    # the case is free again
    r2 = lgk.solve_weightings(cs, W[:2], rho[:2], tol=0.0, max_iter=20)
    assert lgk.fetch_stats(r2)["iters"].tolist() == [20, 20]
