"""Pins for the oracle's LP, simplex and vertex enumeration (CPU only).

Each check ties the oracle to something other than itself: brute-force vertex
enumeration, a closed-form optimum, a library LP solver (HiGHS), strong
duality / KKT conditions, and the primal objective of Sec. 2.A evaluated
directly from doses.
"""
import numpy as np
import pytest
import scipy.optimize

from oracle import kkt as KK
from oracle import lp as L
from oracle import simplex as SX
from oracle import vertex as VX
from synth import cases as SC


def tiny_case(seed, P=4, n_iso=1, S=2, C=1, kinds=(0, 1, 2, 3)):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.05, 1.0, size=(P, n_iso * S * C))
    kind = np.array([kinds[i % len(kinds)] for i in range(P)], np.uint8)
    sid = np.zeros(P, np.uint16)
    lp = L.assemble(phi, kind, sid, n_iso, [20.0], 10.0, 5.0, 3.0, n_sectors=S, n_coll=C)
    return phi, kind, lp


def direct_objective(phi, kind, t, W, n_iso, S, C, d_presc=20.0, d_ld1=10.0,
                     d_ld2=5.0, phi_cal=3.0):
    """Sec. 2.A weighted sum, computed from doses with no reference to A:
    mean target underdose, mean ring / low-dose overdose (relative to their
    threshold), plus w_BOT times the normalised beam-on time."""
    wT, wR, wLD, wBOT = W
    d = phi @ t
    f = 0.0
    for k, D, w, sgn in ((0, d_presc, wT, -1), (1, d_presc, wT, -1), (2, d_presc, wR, 1),
                         (3, d_ld1, wLD, 1), (4, d_ld2, wLD, 1)):
        sel = kind == k
        if sel.any():
            f += w * np.mean(np.maximum(0.0, sgn * (d[sel] / D - 1.0)))
    per_sector = t.reshape(n_iso, S, C).sum(axis=2)
    tau = per_sector.max(axis=1) * phi_cal / d_presc
    return f + wBOT * tau.sum(), tau


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("pre", [False, True])
def test_simplex_equals_vertex_enumeration(seed, pre):
    _, _, lp = tiny_case(seed)
    if pre:
        lp = L.precondition(lp)
    rng = np.random.default_rng(100 + seed)
    W = np.array([[1.0, rng.uniform(0.2, 1), rng.uniform(0, 1), rng.uniform(1e-3, 0.3)]])
    b, _, u = L.bounds(lp, W)
    r = SX.simplex(lp.A, b[:, 0], lp.c, u[:, 0])
    _, vobj, nv = VX.enumerate_vertices(lp.A, b[:, 0], lp.c, u[:, 0])
    assert r.status == "optimal" and nv > 0
    assert abs(r.obj - vobj) <= 1e-10 * max(1.0, abs(vobj))


def test_vertex_enumeration_textbook_lp():
    # min -x1 - x2 s.t. x1 + 2 x2 <= 4, 3 x1 + x2 <= 6, 0 <= x <= 10: optimum at (1.6, 1.2)
    A = np.array([[1.0, 2.0], [3.0, 1.0]])
    x, obj, _ = VX.enumerate_vertices(A, [4.0, 6.0], [-1.0, -1.0], [10.0, 10.0])
    np.testing.assert_allclose(x, [1.6, 1.2], atol=1e-12)
    r = SX.simplex(A, [4.0, 6.0], [-1.0, -1.0], [10.0, 10.0])
    np.testing.assert_allclose(r.x, [1.6, 1.2], atol=1e-12)
    np.testing.assert_allclose(r.lam, [0.4, 0.2], atol=1e-12)   # textbook duals


@pytest.mark.parametrize("phi,wT,wBOT", [(0.5, 1.0, 0.1), (0.5, 1.0, 0.2), (2.0, 0.3, 0.05),
                                         (0.1, 1.0, 0.01)])
def test_one_point_one_beam_closed_form(phi, wT, wBOT):
    """N = 1 isocenter, one sector, one collimator, one target point:
    min w_T (1 - phi t / D)_+ + w_BOT tau, tau >= phi_cal t / D.  Optimum
    min(w_T, w_BOT phi_cal / phi); t* = D/phi if w_T phi > w_BOT phi_cal else 0."""
    D, pc = 20.0, 3.0
    lp = L.assemble(np.array([[phi]]), np.array([0], np.uint8), np.array([0], np.uint16),
                    1, [D], 10.0, 5.0, pc, n_sectors=1, n_coll=1)
    assert lp.A.shape == (2, 2)
    np.testing.assert_allclose(lp.A, [[phi / D, -pc / D], [0.0, 1.0]])
    np.testing.assert_allclose(lp.c, [-1.0, 0.0])
    W = np.array([[wT, 1.0, 0.0, wBOT]])
    b, _, u = L.bounds(lp, W)
    r = SX.simplex(lp.A, b[:, 0], lp.c, u[:, 0])
    best = min(wT, wBOT * pc / phi)
    assert abs(-r.obj - best) <= 1e-14
    t, tau = L.times_from_multipliers(lp, r.lam)
    expect_t = D / phi if wT * phi > wBOT * pc else 0.0
    assert abs(t[0, 0] - expect_t) <= 1e-12 * max(1.0, expect_t)


def test_zero_target_weight_gives_empty_plan():
    _, _, lp = tiny_case(3)
    W = np.array([[0.0, 0.0, 0.0, 0.05]])
    b, _, u = L.bounds(lp, W)
    r = SX.simplex(lp.A, b[:, 0], lp.c, u[:, 0])
    assert abs(r.obj) <= 1e-15
    t, tau = L.times_from_multipliers(lp, r.lam)
    assert np.abs(t).max() <= 1e-14 and np.abs(tau).max() <= 1e-14


@pytest.mark.parametrize("seed", range(4))
def test_assembly_matches_direct_primal_objective(seed):
    """b^T lam + u^T (-(c + A^T lam))_+ with lam = (t, tau) equals the
    Sec. 2.A objective evaluated straight from the doses phi t (pins signs,
    the 1/D scalings, the transposition of phi and the C_S, T blocks)."""
    n_iso, S, C = 2, 3, 2
    phi, kind, lp = tiny_case(seed, P=11, n_iso=n_iso, S=S, C=C, kinds=(0, 1, 2, 3, 4))
    rng = np.random.default_rng(seed)
    W = np.array([1.0, 0.7, 0.4, 0.02])
    t = rng.uniform(0, 30, size=n_iso * S * C)
    f_direct, tau = direct_objective(phi, kind, t, W, n_iso, S, C)
    b, _, u = L.bounds(lp, W[None, :])
    f_lp, viol = KK.planning_objective(lp.A, b[:, 0], lp.c, u[:, 0], np.concatenate([t, tau]))
    assert viol <= 1e-12
    assert abs(f_lp - f_direct) <= 1e-12 * max(1.0, f_direct)


@pytest.fixture(scope="module")
def cfg0():
    case = SC.workload_case(0)
    raw = L.assemble_case(case)
    lp = L.precondition(raw)
    W = SC.slider_weights(3)
    return case, raw, lp, W


def test_workload_shapes():
    expect = {0: (500, 4660), 1: (3750, 41200), 2: (5000, 61600), 3: (8325, 122664)}
    for cfg, (m, n) in expect.items():
        case = SC.workload_case(cfg, with_phi=False)
        assert 25 * case.n_iso == m                       # m = 25 N_iso (Table 1)
        assert case.n_pts + 8 * case.n_iso == n


def test_row_normalisation_invariants(cfg0):
    """Sec. 3.C: after normalising the rows, diag(S) = 2 and |S_ij| <= 1."""
    _, raw, lp, _ = cfg0
    Ar = L.precondition(raw, scale_bot=False).A
    S = Ar @ Ar.T + np.eye(Ar.shape[0])
    np.testing.assert_allclose(np.diag(S), 2.0, atol=1e-13)
    off = S - np.diag(np.diag(S))
    assert np.abs(off).max() <= 1.0 + 1e-13
    assert lp.beta == pytest.approx(4500 / 2000)          # beta formula
    # beta scales only the BOT columns
    np.testing.assert_allclose(lp.A[:, :lp.n_pts], Ar[:, :lp.n_pts], rtol=0, atol=0)
    np.testing.assert_allclose(lp.A[:, lp.n_pts:], lp.beta * Ar[:, lp.n_pts:], rtol=1e-15)


def test_simplex_matches_highs_and_kkt(cfg0):
    """Own simplex = HiGHS (library) on the 3x3 slider grid; KKT residuals and
    strong duality (planning objective at the multipliers = -dual optimum)."""
    _, raw, lp, W = cfg0
    b, _, u = L.bounds(lp, W)
    for j in range(W.shape[0]):
        r = SX.simplex(lp.A, b[:, j], lp.c, u[:, j])
        assert r.status == "optimal"
        bnds = [(0, None if not np.isfinite(x) else x) for x in u[:, j]]
        h = scipy.optimize.linprog(lp.c, A_ub=lp.A, b_ub=b[:, j], bounds=bnds, method="highs")
        # HiGHS stops at its default feasibility tolerance (1e-7); the KKT
        # residuals below certify the simplex optimum to rounding level.
        assert abs(r.obj - h.fun) <= 1e-7 * max(1.0, abs(h.fun))
        k = KK.kkt_residuals(lp.A, b[:, j], lp.c, u[:, j], r.x, r.lam)
        assert k["primal_inf"] <= 1e-9 and k["dual_inf"] <= 1e-9
        assert k["comp"] <= 1e-9 and abs(k["gap"]) <= 1e-9
        f, viol = KK.planning_objective(lp.A, b[:, j], lp.c, u[:, j], r.lam)
        assert viol <= 1e-9 and abs(f + r.obj) <= 1e-9


def test_preprocessing_keeps_optimum(cfg0):
    """Row scaling and the beta column scaling are reformulations: the raw and
    preprocessed LPs have the same optimum, and the recovered sector times give
    the same planning objective on the raw LP."""
    _, raw, lp, W = cfg0
    for j in (0, 4, 8):
        br, _, ur = L.bounds(raw, W[j:j + 1])
        bp, _, up = L.bounds(lp, W[j:j + 1])
        rr = SX.simplex(raw.A, br[:, 0], raw.c, ur[:, 0])
        rp = SX.simplex(lp.A, bp[:, 0], lp.c, up[:, 0])
        assert abs(rr.obj - rp.obj) <= 1e-9 * max(1.0, abs(rr.obj))
        t, tau = L.times_from_multipliers(lp, rp.lam)
        f, viol = KK.planning_objective(raw.A, br[:, 0], raw.c, ur[:, 0],
                                        np.concatenate([t[:, 0], tau[:, 0]]))
        assert viol <= 1e-9 and abs(f + rr.obj) <= 1e-9


def test_rho_rule_and_beta():
    assert L.rho_rule(1e-4, 1e-4, 7.0) == pytest.approx(7.0)
    assert L.rho_rule(1e-2, 1e-4, 7.0) == pytest.approx(0.7)
    assert L.rho_rule(4e-4, 1e-4, rho0=L.RHO0_PAPER) == pytest.approx(1.25e-3)
    lp = L.precondition(tiny_case(0)[2])
    assert L.rho0_for(lp) == pytest.approx(L.RHO0_PER_BETA * lp.beta)


def test_multitarget_bounds():
    """Appendix A multi-target weights: u_kTS = q_kA w_T / N_kTS,
    u_kTI = q_kV w_T / N_kTI, u_kR = (w_R / n) / N_kR."""
    rng = np.random.default_rng(0)
    kind = np.array([0, 0, 1, 2, 0, 1, 1, 2, 2, 3, 4], np.uint8)
    sid = np.array([0, 0, 0, 0, 1, 1, 1, 1, 1, 0, 0], np.uint16)
    phi = rng.uniform(0.1, 1, size=(11, 24))
    lp = L.assemble(phi, kind, sid, 1, [20.0, 20.0], 10.0, 5.0, 3.0,
                    q_area=[0.25, 0.75], q_vol=[0.4, 0.6])
    W = np.array([[2.0, 3.0, 5.0, 0.1]])
    _, _, u = L.bounds(lp, W)
    expect = [0.25 * 2 / 2, 0.25 * 2 / 2, 0.4 * 2 / 1, 1.5 / 1, 0.75 * 2 / 1, 0.6 * 2 / 2,
              0.6 * 2 / 2, 1.5 / 2, 1.5 / 2, 5.0, 5.0]
    np.testing.assert_allclose(u[:11, 0], expect)
    assert np.all(np.isinf(u[11:, 0]))


def test_bf16_round_matches_torch_and_ties():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-45, 30, 20000),
                        [0.0, -0.0, 1.0, 2.0 ** -130, 3.0 * 2.0 ** -135]]).astype(np.float32)
    x = x[np.isfinite(x)]
    ours = L.bf16_round(x.astype(np.float64))
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert L.bf16_round(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert L.bf16_round(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    y = L.bf16_round(rng.standard_normal(1000))
    np.testing.assert_array_equal(L.bf16_round(y), y)   # idempotent
