"""Pins for the oracle ADMM (Eq. admm) and the clinical metrics (CPU only)."""
import numpy as np
import pytest

from oracle import admm as AD
from oracle import lp as L
from oracle import metrics as M
from oracle import simplex as SX
from synth import cases as SC



@pytest.fixture(scope="module")
def cfg0():
    case = SC.workload_case(0)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(3)
    b, l, u = L.bounds(lp, W)
    opt = np.array([SX.simplex(lp.A, b[:, j], lp.c, u[:, j]).obj for j in range(W.shape[0])])
    return case, lp, W, b, l, u, opt


def test_admm_reaches_simplex_optimum_on_small_case():
    """Long run on a small generated case (75 x 384): the ADMM objective
    approaches the simplex optimum.  After 3000 iterations the error is of the
    order of 1 % (as Sec. 3.C reports for its cases); ADMM's tail on LPs is
    slow, so the bound after 60000 iterations is 5e-5 relative."""
    case = SC.make_case([(np.zeros(3), np.full(3, 5.0))], n_target_pts=120, n_ring=80,
                        n_ld1=80, n_ld2=80, n_iso=3, seed=5)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(2)
    b, l, u = L.bounds(lp, W)
    v = np.array([SX.simplex(lp.A, b[:, j], lp.c, u[:, j]).obj for j in range(4)])
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, 2.5e3)   # fixed rho0: this pins convergence, not the rule
    early = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=3000)
    res = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=60000)
    err_early = np.abs(early.objective(lp.c) - v) / np.abs(v)
    err = np.abs(res.objective(lp.c) - v) / np.abs(v)
    assert err_early.max() <= 3e-2
    assert err.max() <= 5e-5 and err.max() < err_early.max() / 100


def test_admm_cfg0_objective_gap_and_invariants(cfg0):
    """rho rule + residual stop at 1e-4: every weighting of the 3x3 grid
    converges and its objective c^T z1 is within 1e-3 of the simplex optimum
    (|obj - obj*| / max(1, |obj*|)); z1 in [l, u], z2 <= b and y2 >= 0 hold
    exactly (projections)."""
    case, lp, W, b, l, u, opt = cfg0
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    res = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=20000, tol=1e-4)
    assert res.converged.all()
    gap = np.abs(res.objective(lp.c) - opt) / np.maximum(1.0, np.abs(opt))
    assert gap.max() <= 1e-3
    assert np.all(res.z1 >= l) and np.all(res.z1 <= u)
    assert np.all(res.z2 <= b)
    assert np.all(res.y2 >= 0.0)
    assert np.all(res.rel_pri <= 1e-4) and np.all(res.rel_dual <= 1e-4)


def test_fixed_iteration_mode_and_column_independence(cfg0):
    case, lp, W, b, l, u, opt = cfg0
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    full = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=40)
    assert np.all(full.iters == 40)
    one = AD.admm(lp.A, lp.c, b[:, 4:5], l[:, 4:5], u[:, 4:5], rho[4:5], max_iter=40)
    np.testing.assert_allclose(one.z1[:, 0], full.z1[:, 4], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(one.y2[:, 0], full.y2[:, 4], rtol=1e-10, atol=1e-14)


def test_q_form_recurrence_equals_literal_admm(cfg0):
    """Algebra the CUDA path relies on.  With q1 = x1 + y1_prev and
    q2 = x2 + y2_prev (so z = P(q), y = q - P(q)):
        rhs = A (2 P1(q1) - q1 - c/rho) + q2 - 2 P2(q2),   v = S^-1 rhs
        q1' = P1(q1) - c/rho - A^T v,                     q2' = v + P2(q2)
    reproduces the literal iterates of Eq. admm."""
    import scipy.linalg
    case, lp, W, b, l, u, opt = cfg0
    A = lp.A
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    n_it = 50
    lit = AD.admm(A, lp.c, b, l, u, rho, max_iter=n_it)
    cf = scipy.linalg.cho_factor(A @ A.T + np.eye(A.shape[0]), lower=True)
    cr = lp.c[:, None] / rho[None, :]
    q1 = np.zeros_like(u)
    q2 = np.zeros_like(b)
    for _ in range(n_it):
        p1 = np.clip(q1, l, u)
        p2 = np.minimum(q2, b)
        v = scipy.linalg.cho_solve(cf, A @ (2 * p1 - q1 - cr) + q2 - 2 * p2)
        q1 = p1 - cr - A.T @ v
        q2 = v + p2
    z1, z2 = np.clip(q1, l, u), np.minimum(q2, b)
    scale = np.abs(lit.y1).max()
    np.testing.assert_allclose(z1, lit.z1, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(q1 - z1, lit.y1, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(z2, lit.z2, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(q2 - z2, lit.y2, rtol=0, atol=1e-12 * scale)


def test_admm_multipliers_give_primal_times(cfg0):
    """Sec. 2.B: rho * y2 approaches the LP multipliers; the sector times it
    gives reach the optimal planning objective within the stop tolerance."""
    from oracle import kkt as KK
    case, lp, W, b, l, u, opt = cfg0
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    res = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=20000, tol=1e-5)
    lam = res.multipliers()
    for j in range(W.shape[0]):
        f, viol = KK.planning_objective(lp.A, b[:, j], lp.c, u[:, j], lam[:, j])
        assert abs(f + opt[j]) <= 2e-3 * abs(opt[j]) + 1e-6
        assert viol <= 1e-3


# ----------------------------------------------------------------- metrics

def _sphere_grid(r_max=14, h=1.0):
    ax = np.arange(-r_max, r_max + h / 2, h)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.sqrt(X ** 2 + Y ** 2 + Z ** 2).ravel()


def test_metrics_analytic_sphere():
    r = _sphere_grid()
    label = np.where(r <= 8.0, 0, -1)
    D = 20.0
    d = np.where(r <= 8.0, D, 0.0)[:, None]
    t = np.zeros((24, 1))
    mt = M.plan_metrics(d, label, [D], t, 1)
    assert mt["coverage"][0] == 1.0 and mt["selectivity"][0] == 1.0 and mt["gi"][0] == 1.0
    # a shell at 60 % of the prescription: GI = voxels within r<=10 / voxels within r<=8
    d2 = np.where(r <= 8.0, D, np.where(r <= 10.0, 0.6 * D, 0.0))[:, None]
    mt2 = M.plan_metrics(d2, label, [D], t, 1)
    assert mt2["gi"][0] == pytest.approx((r <= 10.0).sum() / (r <= 8.0).sum())
    # under-dosing half the target: coverage = that share, selectivity stays 1
    d3 = np.where((r <= 8.0) & (np.arange(r.size) % 2 == 0), D, 0.0)[:, None]
    mt3 = M.plan_metrics(d3, label, [D], t, 1)
    inside = np.flatnonzero(r <= 8.0)
    assert mt3["coverage"][0] == pytest.approx((inside % 2 == 0).mean())
    assert mt3["selectivity"][0] == 1.0


def test_beam_on_time_definition():
    # 2 isocenters, 8 sectors, 3 collimators
    t = np.zeros((2, 8, 3))
    t[0, 2] = [1.0, 2.0, 0.5]      # sector sum 3.5 (longest of iso 0)
    t[0, 5] = [3.0, 0.0, 0.0]
    t[1, 7] = [0.0, 0.0, 4.0]      # longest of iso 1
    t[1, 0] = [1.0, 1.0, 1.0]
    bot = M.beam_on_time(t.reshape(48, 1), 2)
    assert bot[0] == pytest.approx(3.5 + 4.0)


def test_gradient_index_omitted_for_unequal_prescriptions():
    d = np.array([[30.0], [5.0], [25.0]])
    mt = M.plan_metrics(d, np.array([0, -1, 1]), [20.0, 24.0], np.zeros((24, 1)), 1)
    assert np.isnan(mt["gi"][0])
    assert mt["coverage"][0] == 1.0
