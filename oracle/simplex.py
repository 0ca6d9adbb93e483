"""Dense bounded-variable primal simplex for the dual LP (textbook method).

Test infrastructure (see oracle/__init__.py).  The paper's baseline solver is
a dual simplex (Sec. 3.A); the oracle only needs the exact optimum of the
same LP, which any simplex method reaches, so this is the plainest variant:
revised primal simplex with an explicit basis inverse, bound flipping for the
boxed variables, Dantzig pricing and Bland's rule whenever the objective has
stalled (which guarantees termination on degenerate LPs).

Problem:  minimize c^T x  s.t.  A x <= b,  0 <= x <= u  (u may be +inf),
with b >= 0, so x = 0 with slacks s = b is a feasible starting basis.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class SimplexResult:
    x: np.ndarray        # (n,) optimal vertex
    obj: float           # c^T x
    lam: np.ndarray      # (m,) multipliers of A x <= b (>= 0)
    pivots: int
    status: str          # "optimal" | "unbounded" | "iteration_limit"


def simplex(A, b, c, u, *, max_pivots: int = 200000, tol: float = 1e-9,
            feas_tol: float = 1e-10, refactor_every: int = 64,
            stall: int = 30, perturb: float = 1e-8, seed: int = 0) -> SimplexResult:
    A = np.asarray(A, dtype=np.float64)
    b_orig = np.asarray(b, dtype=np.float64).ravel()
    # Degeneracy breaking: most rows have b = 0, which makes the primal simplex
    # stall.  Pivot on b + delta (delta > 0 tiny, random), then evaluate the
    # final (optimal) basis on the original b; reduced costs do not depend on b.
    rng = np.random.Generator(np.random.PCG64(seed))
    b = b_orig + perturb * rng.uniform(0.5, 1.0, size=b_orig.shape)
    c = np.asarray(c, dtype=np.float64).ravel()
    m, n = A.shape
    if np.any(b_orig < 0):
        raise ValueError("simplex start needs b >= 0 (x = 0 feasible)")
    ub = np.concatenate([np.asarray(u, dtype=np.float64).ravel(), np.full(m, np.inf)])
    cost = np.concatenate([c, np.zeros(m)])
    N = n + m

    def col(j):
        if j < n:
            return A[:, j]
        e = np.zeros(m)
        e[j - n] = 1.0
        return e

    basis = np.arange(n, n + m)
    at_upper = np.zeros(N, dtype=bool)      # nonbasic status
    is_basic = np.zeros(N, dtype=bool)
    is_basic[basis] = True
    Binv = np.eye(m)

    def basic_values():
        rhs = b.copy()
        up = np.flatnonzero(at_upper & ~is_basic)
        if up.size:
            struct = up[up < n]
            rhs -= A[:, struct] @ ub[struct]
        return Binv @ rhs

    xB = basic_values()
    obj_prev = np.inf
    stalled = 0
    for piv in range(max_pivots):
        if piv % refactor_every == 0 and piv > 0:
            Bmat = np.column_stack([col(j) for j in basis])
            Binv = np.linalg.inv(Bmat)
            xB = basic_values()
            xB = np.clip(xB, 0.0, ub[basis])
        pi = cost[basis] @ Binv                        # simplex multipliers
        d = cost - np.concatenate([A.T @ pi, pi])      # reduced costs
        eligible = (~is_basic) & (((~at_upper) & (d < -tol)) | (at_upper & (d > tol)))
        cand = np.flatnonzero(eligible)
        if cand.size == 0:
            # Back to the original b.  The basis stays dual feasible (reduced
            # costs do not depend on b); restore primal feasibility with dual
            # simplex pivots (leave the most violated basic variable at its
            # violated bound, enter by the dual ratio test).
            b = b_orig
            for _ in range(10 * m + 100):
                Bmat = np.column_stack([col(j) for j in basis])
                Binv = np.linalg.inv(Bmat)
                xB = basic_values()
                viol = np.maximum(-xB, xB - ub[basis])
                r = int(np.argmax(viol))
                if viol[r] <= 1e-13:
                    break
                below = xB[r] < 0.0
                pi = cost[basis] @ Binv
                d = cost - np.concatenate([A.T @ pi, pi])
                alpha = np.concatenate([Binv[r] @ A, Binv[r]])
                s_dir = -1.0 if below else 1.0   # want x_Br to move by -s_dir
                # x_Br = beta_r - sum alpha_rj x_j: raising x_j changes x_Br by -alpha_rj
                inc = (~is_basic) & (~at_upper) & (s_dir * alpha > tol)
                dec = (~is_basic) & at_upper & (s_dir * alpha < -tol)
                elig = np.flatnonzero(inc | dec)
                if elig.size == 0:
                    return SimplexResult(x=np.full(n, np.nan), obj=np.nan,
                                         lam=np.full(m, np.nan), pivots=piv,
                                         status="infeasible")
                ratio = np.abs(d[elig]) / np.abs(alpha[elig])
                q = int(elig[np.argmin(ratio)])
                jl = basis[r]
                is_basic[jl] = False
                at_upper[jl] = not below
                is_basic[q] = True
                at_upper[q] = False
                basis[r] = q
                piv += 1
            Bmat = np.column_stack([col(j) for j in basis])
            Binv = np.linalg.inv(Bmat)
            xB = np.clip(basic_values(), 0.0, ub[basis])
            pi = np.linalg.solve(Bmat.T, cost[basis])
            x = np.zeros(N)
            x[at_upper & ~is_basic] = ub[at_upper & ~is_basic]
            x[basis] = xB
            return SimplexResult(x=x[:n], obj=float(c @ x[:n]), lam=-pi, pivots=piv,
                                 status="optimal")
        use_bland = stalled >= stall
        q = int(cand[0]) if use_bland else int(cand[np.argmax(np.abs(d[cand]))])
        sigma = 1.0 if not at_upper[q] else -1.0       # +1: increase from 0
        w = Binv @ col(q)
        # ratio test: x_B(t) = x_B - sigma t w, t >= 0
        sw = sigma * w
        t_best, leave, leave_to_upper = ub[q], -1, False   # own bound flip
        piv_tol = max(tol, 1e-7 * float(np.max(np.abs(w))))
        idx = np.flatnonzero(np.abs(sw) > piv_tol)
        if idx.size:
            dec = sw[idx] > 0                          # basic var falls to 0
            ubj = ub[basis[idx]]
            room = np.where(dec, xB[idx], ubj - xB[idx])
            asw = np.abs(sw[idx])
            ok = dec | np.isfinite(ubj)
            # Harris pass 1: largest step with bounds relaxed by feas_tol
            with np.errstate(divide="ignore", invalid="ignore"):
                t_relax = np.where(ok, (np.maximum(room, 0.0) + feas_tol) / asw, np.inf)
                t_exact = np.where(ok, np.maximum(room, 0.0) / asw, np.inf)
            tmin = t_exact.min()
            if tmin < t_best:
                if use_bland:       # exact ties, smallest variable index
                    ties = np.flatnonzero(t_exact <= tmin)
                    pick = ties[np.argmin(basis[idx[ties]])]
                else:               # Harris pass 2: largest pivot magnitude
                    ties = np.flatnonzero(t_exact <= t_relax.min())
                    pick = ties[np.argmax(asw[ties])]
                if t_exact[pick] < t_best:
                    t_best, leave, leave_to_upper = float(t_exact[pick]), int(idx[pick]), bool(~dec[pick])
        if not np.isfinite(t_best):
            return SimplexResult(x=np.full(n, np.nan), obj=-np.inf, lam=np.full(m, np.nan),
                                 pivots=piv, status="unbounded")
        xB = xB - sigma * t_best * w
        xB = np.clip(xB, 0.0, ub[basis])
        if leave < 0:                                  # bound flip, basis unchanged
            at_upper[q] = not at_upper[q]
        else:
            jl = basis[leave]
            enter_val = (ub[q] - t_best) if at_upper[q] else t_best
            is_basic[jl] = False
            at_upper[jl] = leave_to_upper
            is_basic[q] = True
            at_upper[q] = False
            basis[leave] = q
            xB[leave] = enter_val
            # elementary update of the basis inverse
            piv_row = Binv[leave] / w[leave]
            Binv = Binv - np.outer(w, piv_row)
            Binv[leave] = piv_row
        obj = cost[basis] @ xB + cost[at_upper & ~is_basic] @ ub[at_upper & ~is_basic]
        if obj < obj_prev - 1e-12 * max(1.0, abs(obj_prev)):
            stalled = 0
        else:
            stalled += 1
        obj_prev = min(obj, obj_prev)
    return SimplexResult(x=np.full(n, np.nan), obj=np.nan, lam=np.full(m, np.nan),
                         pivots=max_pivots, status="iteration_limit")
