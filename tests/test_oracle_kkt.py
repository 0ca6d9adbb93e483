"""Pins for oracle.kkt.kkt_residuals on a hand-solved LP (CPU only).

    min  -x1 - 2 x2 + x3   s.t.  x1 + x2 - x3 <= 1,   0 <= x1, x2 <= 1,  x3 >= 0 (u = inf)

Worked by hand: x3 buys one unit of room in the row at cost 1, which x1 turns
into a gain of 1, so the optimum is -2 (x* = (0, 1, 0) is one optimal
vertex).  Dual: c + A^T lam = (lam - 1, lam - 2, 1 - lam); the u = inf column
needs 1 - lam >= 0, the others get nu = (1 - lam, 2 - lam) (lam <= 1), so the
dual objective -lam - nu1 - nu2 = lam - 3 is largest at lam* = 1, value -2:
zero duality gap.  Each perturbed point below has a residual worked out by
hand, so a dropped term or a wrong sign in any residual fails a case.
"""
import numpy as np
import pytest

from oracle import kkt as KKT

A = np.array([[1.0, 1.0, -1.0]])
b = np.array([1.0])
c = np.array([-1.0, -2.0, 1.0])
u = np.array([1.0, 1.0, np.inf])


def _k(x, lam):
    return KKT.kkt_residuals(A, b, c, u, np.array(x, dtype=float), np.array([lam], dtype=float))


def test_optimal_pair_has_zero_residuals():
    r = _k([0.0, 1.0, 0.0], 1.0)
    assert r["primal_obj"] == -2.0 and r["dual_obj"] == -2.0
    for key in ("primal_inf", "dual_inf", "comp", "gap"):
        assert r[key] == 0.0, key
    # another optimal primal point (x3 = x1 = 1/2) with the same multiplier
    r = _k([0.5, 1.0, 0.5], 1.0)
    assert r["gap"] == 0.0 and r["primal_inf"] == 0.0 and r["comp"] == 0.0


@pytest.mark.parametrize("x, lam, want", [
    # feasible, suboptimal primal point: c^T x = -1.5, dual -2
    ([0.5, 0.5, 0.0], 1.0, dict(gap=0.5, primal_inf=0.0, dual_inf=0.0, comp=0.0)),
    # suboptimal multiplier: dual objective -0.5 - 0.5 - 1.5 = -2.5
    ([0.0, 1.0, 0.0], 0.5, dict(gap=0.5, primal_inf=0.0, dual_inf=0.0, comp=0.0, dual_obj=-2.5)),
    # row violated by 0.5 (A x = 1.5): |lam * slack| = 0.5
    ([1.0, 1.0, 0.5], 1.0, dict(primal_inf=0.5, comp=0.5, dual_inf=0.0)),
    # upper bound and row violated by 0.25 each
    ([0.0, 1.25, 0.0], 1.0, dict(primal_inf=0.25, comp=0.25)),
    # negative bound
    ([-0.125, 1.0, 0.0], 1.0, dict(primal_inf=0.125)),
    # lam above 1 breaks the u = inf column's reduced cost: nu3 = 0.5
    ([0.0, 1.0, 0.0], 1.5, dict(dual_inf=0.5, primal_inf=0.0)),
    # negative multiplier
    ([0.0, 1.0, 0.0], -0.25, dict(dual_inf=0.25)),
])
def test_perturbed_points(x, lam, want):
    r = _k(x, lam)
    for key, val in want.items():
        assert r[key] == pytest.approx(val, abs=1e-15), (key, r)
