"""Pins for the test-side model of the library's lagged-low-term iteration
(`tests/device_model.py`): it reduces to the literal oracle iteration when
there is no low term or every iteration is full, and it keeps the literal
iteration's fixed points (CPU only)."""
import numpy as np

from oracle import admm as AD
from oracle import lp as L
from synth import cases as SC

from device_model import lagged_admm


def _small_lp():
    case = SC.make_case([(np.zeros(3), np.full(3, 5.0))], n_target_pts=150, n_ring=80, n_ld1=80,
                        n_ld2=80, n_iso=3, seed=17)
    lp = L.precondition(L.assemble_case(case))
    W = SC.slider_weights(2)
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, 2.5e3)
    return lp, b, l, u, rho


def test_lagged_low_term_reduces_to_literal():
    """With A_hi = A (no low term) or a refresh every iteration, the lagged
    iteration is the literal one, step for step."""
    lp, b, l, u, rho = _small_lp()
    ref = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=40)
    for hi, refresh in ((lp.A, 10), (L.bf16_round(lp.A), 1)):
        got = lagged_admm(lp.A, hi, lp.c, b, l, u, rho, max_iter=40, refresh=refresh, restart=50)
        np.testing.assert_allclose(got.z1, ref.z1, rtol=0, atol=1e-13)
        np.testing.assert_allclose(got.y2, ref.y2, rtol=0, atol=1e-13)


def test_lagged_low_term_keeps_the_fixed_point():
    """The lagged iteration differs along the way but has the literal
    iteration's fixed points: after the same (large) number of iterations
    both sit at the same objective, and from a nearly converged literal state
    a run of lagged steps stays where the literal steps stay."""
    lp, b, l, u, rho = _small_lp()
    hi = L.bf16_round(lp.A)
    lit = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=20000)
    lag = lagged_admm(lp.A, hi, lp.c, b, l, u, rho, max_iter=20000, refresh=10, restart=50)
    np.testing.assert_allclose(lag.objective(lp.c), lit.objective(lp.c), rtol=0, atol=2e-6)
    st = (lit.z1, lit.z2, lit.y1, lit.y2)
    a = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=30, state=st)
    c = lagged_admm(lp.A, hi, lp.c, b, l, u, rho, max_iter=30, refresh=10, restart=50, state=st)
    drift = np.abs(a.z1 - lit.z1).max() + np.abs(a.y2 - lit.y2).max()
    assert np.abs(c.z1 - a.z1).max() + np.abs(c.y2 - a.y2).max() <= 10 * drift + 1e-12
    # along the way the light steps do differ from the literal ones
    a = AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=5)
    c = lagged_admm(lp.A, hi, lp.c, b, l, u, rho, max_iter=5, refresh=10, restart=50)
    assert np.abs(a.z1 - c.z1).max() > 0
