"""Organ-at-risk maximum doses (Appendix A: OAR points are columns with
c = +1 and no upper bound, i.e. hard constraints d_O <= D_O of the primal
plan) in the oracle.  A maximum dose at 60 % of what the unconstrained plan
gives must bind: the simplex plan meets it exactly, the planning objective
gets worse, and the FP64 ADMM at tol 1e-4 approaches the same optimum."""
import numpy as np
import pytest

from oracle import admm as AD
from oracle import lp as L
from oracle import simplex as SX
from synth import cases as SC

TARGETS = [(np.zeros(3), np.full(3, 6.0))]
BASE = dict(n_target_pts=200, n_ring=100, n_ld1=100, n_ld2=100, n_iso=4, seed=5)
OAR = ((10.0, 0.0, 0.0), (2.5, 2.5, 2.5))
W = np.array([[1.0, 1.0, 0.5, 1e-4], [1.0, 1.0, 0.5, 1e-3]])


def _solve(case):
    lp = L.precondition(L.assemble_case(case))
    b, l, u = L.bounds(lp, W)
    res = [SX.simplex(lp.A, b[:, j], lp.c, u[:, j]) for j in range(W.shape[0])]
    oar = case.kind == SC.KIND_OAR
    dmax = []
    for r in res:
        t, _ = L.times_from_multipliers(lp, r.lam)
        dmax.append((case.phi[oar] @ t[:, 0]).max())
    return lp, b, l, u, np.array([r.obj for r in res]), np.array(dmax)


@pytest.fixture(scope="module")
def cases():
    free = SC.make_case(TARGETS, **BASE, oars=[OAR + (1e9,)], n_oar=40)
    _, _, _, _, obj_free, d_free = _solve(free)
    d_o = 0.6 * d_free.min()
    con = SC.make_case(TARGETS, **BASE, oars=[OAR + (d_o,)], n_oar=40)
    return dict(free=free, obj_free=obj_free, d_free=d_free, con=con, d_o=d_o)


def test_generator_oar_points(cases):
    con = cases["con"]
    oar = con.kind == SC.KIND_OAR
    assert oar.sum() == 40 and np.all(con.struct_id[oar] == 0)
    assert np.all(np.linalg.norm(con.points[oar] - np.array(OAR[0]), axis=1) <= 2.5 + 1.0)
    assert con.d_oar.shape == (1,) and con.d_oar[0] == pytest.approx(cases["d_o"])
    # the other classes are drawn exactly as without organs at risk
    plain = SC.make_case(TARGETS, **BASE)
    np.testing.assert_array_equal(con.points[~oar], plain.points)


def test_oar_maximum_dose_binds_at_the_simplex_optimum(cases):
    lp, b, l, u, obj, dmax = _solve(cases["con"])
    d_o = cases["d_o"]
    assert np.all(dmax <= d_o * (1 + 1e-9))
    assert np.all(dmax >= d_o * (1 - 1e-6))           # active
    # a hard constraint can only make the plan worse: the dual optimum drops
    assert np.all(obj < cases["obj_free"] - 1e-3)
    # and the unconstrained plans do exceed the limit
    assert np.all(cases["d_free"] > d_o)


def test_admm_reaches_the_constrained_optimum(cases):
    con = cases["con"]
    lp, b, l, u, obj, _ = _solve(con)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    ref = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=60000, tol=1e-4)
    assert ref.converged.all()
    gap = np.abs(ref.objective(lp.c) - obj) / np.maximum(1.0, np.abs(obj))
    assert gap.max() <= 1e-3
    t, _ = L.times_from_multipliers(lp, ref.multipliers())
    dmax = (con.phi[con.kind == SC.KIND_OAR] @ t).max(axis=0)
    assert np.all(dmax <= cases["d_o"] * 1.005)
