"""GPU parity of the solve refinement (lgk_params.solve_refine).

The x-step of Eq. admm (Sec. 2.B, Eq. partial_elimination) solves S v = rhs
with S = A A^T + I and then sets x1 = r1 - A^T v, x2 = v + w, so the split's
constraint holds up to the solve's residual: A x1 - x2 = rhs - S v.  The
library multiplies by an explicit S^{-1} held as three BF16 terms with FP32
sums; when rhs lies along the directions S magnifies, v is ~10^3 times
smaller than rhs and those sums lose the accuracy of v.  A refinement step
computes e = rhs - S v (S as three BF16 terms) and adds S^{-1} e.

The test case has few isocenters and many points (A 500 x 60160, beta = 30):
S is as ill-conditioned as on the large cases while the FP64 oracle stays
cheap.  From a common state after 300 oracle iterations, one device
iteration with 0, 1 and 2 refinement steps: the constraint residual
||rhs - S v|| / ||rhs|| of the device's v (evaluated by the oracle in FP64 on
the two-term matrix) must fall with each step, and the state must agree with
the oracle's iteration element by element within the one-step bound of
tests/test_gpu_parity.py.  Then converged plans with refinement on the 9
weightings of the sphere case meet the same gates as without it.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import admm as AD
from oracle import lp as L
from oracle import simplex as SX
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


def make(lgk, case, **kw):
    return lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                           case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                           params=lgk.default_params(**kw))


def two_term(A):
    hi = L.bf16_round(A)
    return hi + L.bf16_round(A - hi)


def test_refinement_shrinks_the_solve_residual(lgk):
    case = SC.make_case([(np.zeros(3), np.full(3, 10.0))], n_target_pts=18000, n_ring=14000,
                        n_ld1=14000, n_ld2=14000, n_iso=20, seed=71)
    lp = L.precondition(L.assemble_case(case))
    assert lp.m == 500 and abs(lp.beta - 30.0) < 1e-12
    g = SC.slider_weights(3)
    W = g[[0, 2, 4]]
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    A = two_term(lp.A)
    o = AD.admm(A, lp.c, b, l, u, rho, max_iter=300)
    q1, q2 = (o.z1 + o.y1).T, (o.z2 + o.y2).T
    S = A @ A.T + np.eye(lp.m)
    chol = scipy.linalg.cho_factor(S, lower=True)
    # the exact iteration from that state
    z1, z2 = np.clip(q1.T, l, u), np.minimum(q2.T, b)
    rhs = A @ (2 * z1 - q1.T - lp.c[:, None] / rho[None, :]) + q2.T - 2 * z2
    ref = AD.admm(A, lp.c, b, l, u, rho, max_iter=1, state=(o.z1, o.z2, o.y1, o.y2))
    r1, r2 = ref.z1 + ref.y1, ref.z2 + ref.y2
    bound = np.linalg.norm(A, 2) ** 2 * 2.0 ** -17
    resid = []
    for steps in (0, 1, 2):
        cs = make(lgk, case, lo_refresh=0, solve_refine=steps)
        res = lgk.solve_weightings_warm(cs, W, rho, q1_init=q1, q2_init=q2, tol=0.0, max_iter=1)
        g1, g2 = lgk.fetch_state(res)
        v = g2.T - z2                                       # q2' = v + P2(q2)
        resid.append(np.linalg.norm(rhs - S @ v, axis=0) / np.linalg.norm(rhs, axis=0))
        assert np.abs(g1.T - r1).max() <= bound * np.abs(r1).max(), steps
        assert np.abs(g2.T - r2).max() <= bound * np.abs(r2).max(), steps
        cs.close()
    ratio = np.linalg.norm(np.abs(scipy.linalg.cho_solve(chol, np.eye(lp.m))) @ np.abs(rhs), axis=0) \
        / np.linalg.norm(scipy.linalg.cho_solve(chol, rhs), axis=0)
    assert ratio.min() > 30, ratio                        # the cancellation this case is built for
    assert np.all(resid[1] < 0.5 * resid[0]), resid
    assert np.all(resid[2] <= resid[1] * 1.5), resid
    assert resid[2].max() < 1e-4, resid


def test_converged_parity_with_refinement(lgk):
    case = SC.workload_case(0)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(3)
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    opt = np.array([SX.simplex(lp.A, b[:, j], lp.c, u[:, j]).obj for j in range(W.shape[0])])
    cs = make(lgk, case, solve_refine=1)
    res = lgk.solve_weightings(cs, W, rho, tol=5e-5, max_iter=20000)     # 1e-3 objective bar headroom
    st = lgk.fetch_stats(res)
    assert st["converged"].all()
    gap = np.abs(st["obj"] - opt) / np.maximum(1.0, np.abs(opt))
    assert gap.max() <= 1e-3, gap
    assert st["rel_pri"].max() <= 1e-4 and st["rel_dual"].max() <= 1e-4
    ck = lgk.fetch_check(res)
    assert np.all(ck["primal"] <= 1e-4), ck["primal"]    # refined: within tol itself
    # the profile shows the refinement's launches: 2 solves per iteration
    cs_p = make(lgk, case, solve_refine=1, profile=1)
    p = lgk.fetch_profile(lgk.solve_weightings(cs_p, W, rho, tol=0.0, max_iter=20))
    assert p["solve"][1] == 40 and p["sv"][1] == 20 and p["reduce_err"][1] == 20


def test_refinement_switched_on_mid_solve(lgk):
    """refine_after: a solve still running after that many iterations
    continues with one refinement step per iteration (re-captured graph, same
    state); the plans meet the gates of the refined solve, and the profile
    counts the refinement's launches only after the switch."""
    case = SC.workload_case(0)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(3)
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    opt = np.array([SX.simplex(lp.A, b[:, j], lp.c, u[:, j]).obj for j in range(W.shape[0])])
    cs = make(lgk, case, refine_after=200, profile=1)
    res = lgk.solve_weightings(cs, W, rho, tol=5e-5, max_iter=20000)
    st = lgk.fetch_stats(res)
    assert st["converged"].all() and st["iters"].max() > 250
    gap = np.abs(st["obj"] - opt) / np.maximum(1.0, np.abs(opt))
    assert gap.max() <= 1e-3, gap
    assert np.all(lgk.fetch_check(res)["primal"] <= 1e-4)
    p = lgk.fetch_profile(res)
    n_it = p["gemm1"][1]
    assert n_it == st["iters"].max()
    assert p["sv"][1] == n_it - 200 and p["reduce_err"][1] == p["sv"][1]
    assert p["solve"][1] == n_it + p["sv"][1]
    # refine_after = 0: never
    cs0 = make(lgk, case, refine_after=0, profile=1)
    p0 = lgk.fetch_profile(lgk.solve_weightings(cs0, W, rho, tol=0.0, max_iter=300))
    assert p0["sv"][1] == 0 and p0["solve"][1] == 300
