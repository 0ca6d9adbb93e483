"""GPU parity of the plan check (lgk_fetch_check, and the same check inside
lgk_solve_stream) against the oracle.

The device evaluates each finished plan in FP64 against its exact LP
(Sec. 2.B: the plan is the scaled multipliers rho y2; Eq. dual_problem with
the bounds of Appendix A).  Here the oracle evaluates the same quantities
from the same device state (fetch_state), with its own code:
oracle.kkt.planning_objective for the weighted-sum objective of Sec. 2.A and
the hard-constraint violation, plain numpy for the rest, on the matrix the
form iterates on.  Both sides are FP64 sums of the same terms in different
orders (the tolerances, per product path, are stated at TOLS below).
Converged plans of the 9-weighting sphere case then pass the primal check
the benchmark counts a plan by (||(A z1 - b)_+|| <= 2 tol (1 + ||A||_2)
||z||), with FP64 duality gaps of the order of the 1e-3 objective bar (the
gap of a plan stopped at relative residual 1e-4 is not bounded by 1e-3: it
adds both sides' distances to the optimum).
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
    out = {k: np.empty(K) for k in ("obj", "plan", "gap", "infeas", "hard", "bound", "primal")}
    a_norm = np.linalg.norm(A, 2)
    z2 = np.minimum(q2.T, b32)
    for j in range(K):
        obj = float(lp.c @ z1[:, j])
        plan, viol = KK.planning_objective(A, b[:, j], lp.c, u[:, j], lam[:, j])
        Az = A @ z1[:, j]
        fin = np.isfinite(u[:, j])
        out["obj"][j] = obj
        out["plan"][j] = plan
        out["gap"][j] = (obj + plan) / max(1.0, abs(obj))
        out["infeas"][j] = np.linalg.norm(np.maximum(Az - b[:, j], 0.0)) / np.linalg.norm(b[:, j])
        out["hard"][j] = viol / lam[:, j].max()
        out["bound"][j] = max(0.0, float(np.max(z1[fin, j] - u[fin, j])))
        zn = np.sqrt(np.sum(z1[:, j] ** 2) + np.sum(z2[:, j] ** 2))
        out["primal"][j] = np.linalg.norm(np.maximum(Az - b[:, j], 0.0)) / ((1 + a_norm) * zn)
    return out


# tolerances of the check against the oracle (same state, same matrix):
#   FP64 products (the FP32 form, or check_fp64 = 1): FP64 sums in another
#   order, 1e-9 (primal: the power-iteration ||A||_2, 1e-3);
#   tensor-core products (the two-term form's default): exact products, FP32
#   sums over 64 columns, FP64 across them; measured against the oracle on the
#   sphere case: plan 1.5e-6, gap 5e-4 of its (small) value, infeas and
#   primal 5.3e-3, hard 6.3e-4 (relative), each allowed ~5x.
TOLS = {"fp64": dict(plan=1e-9, gap=1e-9, infeas=1e-5, hard=1e-9, primal=1e-3),
        "tc": dict(plan=1e-5, gap=1e-6, infeas=3e-2, hard=3e-3, primal=3e-2)}


@pytest.mark.parametrize("prec, fp64", [(0, 0), (2, 1), (2, 0)],
                         ids=["fp32", "bf16x3_fp64_products", "bf16x3_tensor_cores"])
def test_check_matches_oracle_and_gates(lgk, cfg0, prec, fp64):
    c = cfg0
    lp = c["lp"]
    cs = make(lgk, c["case"], prec, check_fp64=fp64)
    A = lp_matrix(lp, lgk, prec)
    res = lgk.solve_weightings(cs, c["W"], c["rho"], tol=TOL, max_iter=20000)
    st = lgk.fetch_stats(res)
    assert st["converged"].all()
    chk = lgk.fetch_check(res)
    q1, q2 = lgk.fetch_state(res)
    ref = oracle_check(lp, A, c["b"], c["u"], c["W"], c["rho"], q1, q2)
    t = TOLS["tc" if prec == 2 and not fp64 else "fp64"]
    scale = np.abs(lp.c) @ np.abs(np.clip(q1.T, 0, c["u"]))    # c^T z1 sums terms of both signs
    np.testing.assert_allclose(chk["obj"], ref["obj"], rtol=0, atol=1e-12 * scale.max())
    np.testing.assert_allclose(chk["obj"], st["obj"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(chk["plan"], ref["plan"], rtol=t["plan"])
    np.testing.assert_allclose(chk["gap"], ref["gap"], rtol=0, atol=t["gap"])
    np.testing.assert_allclose(chk["infeas"], ref["infeas"], rtol=t["infeas"])
    np.testing.assert_allclose(chk["hard"], ref["hard"], rtol=t["hard"], atol=1e-12)
    np.testing.assert_allclose(chk["bound"], ref["bound"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(chk["primal"], ref["primal"], rtol=t["primal"])
    # the plans that stopped at relative residual 1e-4 pass the primal check
    # the benchmark counts a plan by (<= 2 tol: the stop's bound plus an
    # x-step solve error of up to the same size), and their FP64 duality gaps
    # are of the order of the objective bar
    assert np.all(chk["primal"] <= 2 * TOL), chk["primal"]
    assert np.all(np.abs(chk["gap"]) <= 3e-3), chk["gap"]


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
    for k in ("obj", "plan", "gap", "infeas", "hard", "bound", "primal"):
        np.testing.assert_allclose(s["check"][k][:4], batch[k][:4], rtol=1e-9, atol=1e-15, err_msg=k)
    assert np.isfinite(s["check"]["plan"]).all()
