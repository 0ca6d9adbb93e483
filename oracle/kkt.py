"""Optimality checks and the planning objective (Sec. 2.A, Appendix A).

Test infrastructure (see oracle/__init__.py).

The dual LP  min c^T x,  A x <= b,  0 <= x <= u  has the Lagrange dual
    max  -b^T lam - u^T nu   s.t.  c + A^T lam + nu >= 0,  lam, nu >= 0,
and for a given lam the best nu is (-(c + A^T lam))_+ .  With lam = the sector
times and isocenter beam-on times (Sec. 2.B: the primal solution is rho y*),
b^T lam + u^T nu is exactly the weighted-sum objective of Sec. 2.A: the mean
underdose of the target points, the mean overdose of ring and low-dose points,
and w_BOT times the (normalised) beam-on time; the u = inf columns (OAR points
and the BOT coupling) turn into the hard constraints  d_O <= D_O  and
tau_i >= C_S t restricted to isocenter i.
"""
from __future__ import annotations

import numpy as np


def planning_objective(A, b, c, u, lam, *, tol: float = 1e-9):
    """Weighted-sum objective of Sec. 2.A at multipliers lam, and the largest
    violation of the hard constraints (u = inf columns).  Returns (obj, viol)."""
    lam = np.asarray(lam, dtype=np.float64)
    g = -(np.asarray(c) + A.T @ lam)         # g_j > 0 : hinge active
    fin = np.isfinite(u)
    obj = float(b @ lam + np.sum(u[fin] * np.maximum(g[fin], 0.0)))
    viol = float(np.max(g[~fin], initial=0.0))
    return obj, max(viol, 0.0)


def kkt_residuals(A, b, c, u, x, lam):
    """Scaled KKT residuals of (x, lam) for  min c^T x, Ax <= b, 0 <= x <= u:
    primal infeasibility, dual infeasibility (lam < 0), complementary slackness
    of the rows, and the duality gap c^T x - (-b^T lam - u^T nu)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    slack = b - A @ x
    p_inf = max(float(np.max(-slack, initial=0.0)), float(np.max(-x, initial=0.0)),
                float(np.max((x - u)[np.isfinite(u)], initial=0.0)))
    d_inf = float(np.max(-lam, initial=0.0))
    g = np.asarray(c) + A.T @ lam            # reduced costs
    nu = np.maximum(-g, 0.0)
    fin = np.isfinite(u)
    d_inf = max(d_inf, float(np.max(nu[~fin], initial=0.0)))
    comp = float(np.max(np.abs(lam * slack), initial=0.0))
    dual_obj = -float(b @ lam) - float(u[fin] @ nu[fin])
    gap = float(c @ x) - dual_obj
    return dict(primal_inf=p_inf, dual_inf=d_inf, comp=comp, gap=gap,
                primal_obj=float(c @ x), dual_obj=dual_obj)
