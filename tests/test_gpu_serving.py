"""Serving loop (lgk_server): admission under a device-memory budget, requests
overlapping on the device, and results that are the same alone and in the mix
(bitwise: every reduction of the solve has a fixed order)."""
import numpy as np
import pytest

from synth import cases as SC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk as mod
    return mod


def small_case(seed, n_iso):
    rng = np.random.default_rng(seed)
    r = float(rng.uniform(5.0, 9.0))
    return SC.make_case([(np.zeros(3), np.full(3, r))], n_target_pts=int(rng.integers(400, 900)),
                        n_ring=300, n_ld1=300, n_ld2=300, n_iso=n_iso, seed=seed)


def submit(server, case, W):
    return server.submit(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                         case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal, W)


def test_result_is_the_same_alone_and_in_the_mix(lgk):
    W = SC.slider_weights(3)
    target = small_case(11, 12)
    alone = lgk.Server(workers=1, tol=1e-4)
    rid = submit(alone, target, W)
    info_a, t_a, tau_a = alone.wait(rid, target.n_iso, W.shape[0])
    alone.close()
    assert info_a["status"] == 0 and info_a["converged"] == 9
    mix = lgk.Server(workers=3, tol=1e-4)
    others = [small_case(20 + k, 8 + 2 * k) for k in range(5)]
    ids = [submit(mix, others[0], W), submit(mix, others[1], W), submit(mix, target, W)]
    ids += [submit(mix, c, W) for c in others[2:]]
    got = {}
    for k, rid in enumerate(ids):
        case = target if k == 2 else others[k if k < 2 else k - 1]
        got[rid] = mix.wait(rid, case.n_iso, W.shape[0])
    mix.close()
    info_m, t_m, tau_m = got[ids[2]]
    assert info_m["status"] == 0
    np.testing.assert_array_equal(t_m, t_a)
    np.testing.assert_array_equal(tau_m, tau_a)
    assert all(v[0]["status"] == 0 for v in got.values())
    # the times come back in the order of the input weightings: sector times >= 0
    assert np.all(t_m >= 0)


def test_admission_budget(lgk):
    W = SC.slider_weights(2)
    c = small_case(31, 10)
    # a budget too small for any request: refused at submit, nothing queued
    tiny = lgk.Server(workers=2, hbm_budget=1 << 20)
    with pytest.raises(lgk.LgkError) as e:
        submit(tiny, c, W)
    assert e.value.code == 3
    tiny.close()
    # a budget for about one request at a time: all complete, FIFO order
    probe = lgk.Server(workers=1)
    rid = submit(probe, c, W)
    info, _, _ = probe.wait(rid, c.n_iso, 4)
    probe.close()
    one = lgk.Server(workers=3, hbm_budget=int(info["footprint"] * 1.5))
    ids = [submit(one, c, W) for _ in range(4)]
    infos = [one.wait(i, c.n_iso, 4)[0] for i in ids]
    one.close()
    assert all(i["status"] == 0 for i in infos)
    # with room for one request, they ran one after another: each waited for
    # the previous (queue time grows)
    q = [i["queue_ms"] for i in infos]
    assert q[3] > q[0]


def test_request_joins_a_running_stream_and_matches_alone(lgk):
    """Continuous batching: a resident case (lgk_server_open) runs one
    streaming solve of 8 columns; a 9-weighting request submitted while a
    25-weighting request of the same case is on the GPU joins that stream
    (its first weighting takes a column before the other request is done).
    Its plans equal those of the same request served alone, bit for bit:
    columns never interact and every column starts the same way."""
    import time
    case = small_case(41, 12)
    W9, W25 = SC.slider_weights(3), SC.slider_weights(5)
    args = (case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area, case.q_vol,
            case.d_ld1, case.d_ld2, case.phi_cal)
    alone = lgk.Server(workers=1, tol=1e-4, stream_width=8)
    cid = alone.open(*args)
    rid = alone.submit_to(cid, W9)
    info_a, t_a, tau_a = alone.wait(rid, case.n_iso, 9)
    alone.close_case(cid)
    alone.close()
    assert info_a["status"] == 0 and info_a["converged"] == 9

    mix = lgk.Server(workers=1, tol=1e-4, stream_width=8)
    cid = mix.open(*args)
    t0 = time.perf_counter()
    big = mix.submit_to(cid, W25)
    time.sleep(0.05)
    t1 = time.perf_counter()
    rid = mix.submit_to(cid, W9)
    info_m, t_m, tau_m = mix.wait(rid, case.n_iso, 9)
    info_b, _, _ = mix.wait(big, case.n_iso, 25)
    mix.close_case(cid)
    mix.close()
    assert info_m["status"] == 0 and info_b["status"] == 0
    assert info_m["converged"] == 9 and info_b["converged"] == 25
    # the 9-weighting request started while the 25-weighting one was running
    start_9 = (t1 - t0) * 1e3 + info_m["queue_ms"]
    assert start_9 < info_b["total_ms"], (start_9, info_b["total_ms"])
    np.testing.assert_array_equal(t_m, t_a)
    np.testing.assert_array_equal(tau_m, tau_a)
    assert info_m["max_iters"] == info_a["max_iters"]


def test_closed_case_refuses_requests(lgk):
    case = small_case(43, 10)
    srv = lgk.Server(workers=1, tol=1e-4, stream_width=8)
    cid = srv.open(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                   case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal)
    rid = srv.submit_to(cid, SC.slider_weights(2))
    srv.close_case(cid)
    with pytest.raises(lgk.LgkError) as e:
        srv.submit_to(cid, SC.slider_weights(2))
    assert e.value.code == 1
    info, _, _ = srv.wait(rid, case.n_iso, 4)
    assert info["status"] == 0 and info["converged"] == 4
    srv.close()
