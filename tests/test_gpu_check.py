"""GPU parity of the FP64 plan check (lgk_fetch_check, and the same check
inside lgk_solve_stream) against the oracle.

The device evaluates each finished plan in FP64 against its exact LP
(Sec. 2.B: the plan is the scaled multipliers rho y2; Eq. dual_problem with
the bounds of Appendix A).  Here the oracle evaluates the same quantities
from the same device state (fetch_state), with its own code:
oracle.kkt.planning_objective for the weighted-sum objective of Sec. 2.A and
the hard-constraint violation, plain numpy for the rest, on the matrix the
form iterates on.  Both sides are FP64 sums of the same terms in different
orders: relative agreement 1e-9 (the |A| z1 scale of the infeasibility is an
FP32 sum on the device: 1e-5).  Converged plans of the 9-weighting sphere case
then meet the gates the benchmark counts a plan by: duality gap <= 1e-3 and
backward-error infeasibility <= 1e-4.
"""
import numpy as np
import pytest

from oracle import kkt as KK
from oracle import lp as L
from synth import cases as SC

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lgk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk as mod
    return mod


@pytest.fixture(scope="module")
def cfg0():
    case = SC.workload_case(0)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(3)
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    return dict(case=case, lp=lp, W=W, b=b, l=l, u=u, rho=rho)


def make(lgk, case, prec, **kw):
    return lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                           case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                           params=lgk.default_params(precision=prec, **kw))


def lp_matrix(lp, lgk, prec):
    if prec == lgk.PREC_FP32:
        return lp.A.astype(np.float32).astype(np.float64)
    hi = L.bf16_round(lp.A)
    return hi + L.bf16_round(lp.A - hi)


def oracle_check(lp, A, b, u, W, rho, q1, q2):
    """The check's quantities from a device state, by the oracle.  The plan
    is the device's: z1 clipped to the FP32 bounds, lam from the FP32 b and
    rho the iteration used."""
    f32 = lambda x: np.asarray(x, dtype=np.float32).astype(np.float64)
    K = W.shape[0]
    u32 = f32(u)
    b32 = np.zeros_like(b)
    b32[lp.n_beams:] = f32(f32(W[:, 3])[None, :] * lp.row_scale[lp.n_beams:, None])
    z1 = np.clip(q1.T, 0.0, u32)
    lam = f32(rho)[None, :] * np.maximum(q2.T - b32, 0.0)
    out = {k: np.empty(K) for k in ("obj", "plan", "gap", "infeas", "hard", "bound")}
    for j in range(K):
        obj = float(lp.c @ z1[:, j])
        plan, viol = KK.planning_objective(A, b[:, j], lp.c, u[:, j], lam[:, j])
        Az = A @ z1[:, j]
        fin = np.isfinite(u[:, j])
        out["obj"][j] = obj
        out["plan"][j] = plan
        out["gap"][j] = (obj + plan) / max(1.0, abs(obj))
        out["infeas"][j] = (np.linalg.norm(np.maximum(Az - b[:, j], 0.0))
                            / np.linalg.norm(np.abs(A) @ z1[:, j]))
        out["hard"][j] = viol / lam[:, j].max()
        out["bound"][j] = max(0.0, float(np.max(z1[fin, j] - u[fin, j])))
    return out


@pytest.mark.parametrize("prec", [0, 2], ids=["fp32", "bf16x3"])
def test_check_matches_oracle_and_gates(lgk, cfg0, prec):
    c = cfg0
    lp = c["lp"]
    cs = make(lgk, c["case"], prec)
    A = lp_matrix(lp, lgk, prec)
    res = lgk.solve_weightings(cs, c["W"], c["rho"], tol=TOL, max_iter=20000)
    st = lgk.fetch_stats(res)
    assert st["converged"].all()
    chk = lgk.fetch_check(res)
    q1, q2 = lgk.fetch_state(res)
    ref = oracle_check(lp, A, c["b"], c["u"], c["W"], c["rho"], q1, q2)
    scale = np.abs(lp.c) @ np.abs(np.clip(q1.T, 0, c["u"]))    # c^T z1 sums terms of both signs
    np.testing.assert_allclose(chk["obj"], ref["obj"], rtol=0, atol=1e-12 * scale.max())
    np.testing.assert_allclose(chk["obj"], st["obj"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(chk["plan"], ref["plan"], rtol=1e-9)
    np.testing.assert_allclose(chk["gap"], ref["gap"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(chk["infeas"], ref["infeas"], rtol=1e-5)
    np.testing.assert_allclose(chk["hard"], ref["hard"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(chk["bound"], ref["bound"], rtol=0, atol=1e-15)
    # the plans that stopped at relative residual 1e-4 meet the LP gates
    assert np.all(np.abs(chk["gap"]) <= 1e-3), chk["gap"]
    assert np.all(chk["infeas"] <= TOL), chk["infeas"]


def test_check_inside_the_stream_matches_fetch_check(lgk, cfg0):
    """The stream runs the same check on each weighting's column when it
    stops: the 9 weightings through 4 columns, each checked before its column
    is refilled, equal fetch_check of a 9-column batch of the same fixed
    iteration count (columns never interact)."""
    c = cfg0
    cs = make(lgk, c["case"], 2)
    n = 50
    s = lgk.solve_stream(cs, c["W"], c["rho"], tol=0.0, max_iter=n, width=4, check=True)
    batch = lgk.fetch_check(lgk.solve_weightings(cs, c["W"], c["rho"], tol=0.0, max_iter=n))
    for k in ("obj", "plan", "gap", "infeas", "hard", "bound"):
        np.testing.assert_allclose(s["check"][k][:4], batch[k][:4], rtol=1e-9, atol=1e-15, err_msg=k)
    assert np.isfinite(s["check"]["plan"]).all()
