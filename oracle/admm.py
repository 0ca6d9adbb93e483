"""Literal scaled-form ADMM on the dual LP, batched over weightings (Sec. 2.B).

Test infrastructure (see oracle/__init__.py).  Plain FP64 numpy; the linear
solve with S = A A^T + I uses a library Cholesky factorisation.

Splitting of Eq. dual_problem_admm: x = (x1, x2) in the affine set
{A x1 = x2}, copies z = (z1, z2) with z1 in [l, u] and z2 <= b.  One iteration
(Eq. admm), with the x-step replaced by its closed form (Eq. partial_elimination
and the x-update that follows it):

    r1   = z1 - y1 - c / rho
    v    = S^{-1} (A r1 - z2 + y2)             S = A A^T + I
    x1   = r1 - A^T v
    x2   = v + z2 - y2
    z1'  = clip(x1 + y1, l, u)
    z2'  = min(x2 + y2, b)
    y1'  = y1 + x1 - z1'
    y2'  = y2 + x2 - z2'

All quantities are matrices whose K columns are the weightings (end of
Sec. 2.B); rho is a per-column vector (Sec. 3.C allows a distinct rho per
weighting because rho only enters through the iterates).

Stopping (the paper runs a fixed iteration count, Sec. 3.D; this reading adds
the residual test of Boyd et al., Sec. 3.3 of their monograph): with
r = x' - z' and s = rho (z' - z), column j stops once
    ||r|| <= eps_abs sqrt(n+m) + tol max(||x'||, ||z'||)   and
    ||s|| <= eps_abs sqrt(n+m) + tol ||rho y'||,
checked every `check_every` iterations; a stopped column keeps its iterate.

Per-column penalty adaptation (`balance`, optional; not in the paper, which
fixes rho per weighting by Eq. rho_rule): residual balancing (Boyd et al.,
Sec. 3.4.1 of their monograph) applied per column every `every` iterations
(a multiple of check_every, so the residuals of that iteration's test are
used): if rel_pri > mu rel_dual then rho <- tau rho, if rel_dual > mu rel_pri
then rho <- rho / tau, at most `max_changes` times per column.  S = A A^T + I
does not depend on rho (Sec. 2.B), so a change costs only the rescaling of
the scaled dual variables, y <- y rho_old / rho_new, which keeps the
unscaled multipliers rho y.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg


@dataclasses.dataclass
class AdmmResult:
    z1: np.ndarray      # (n, K)
    z2: np.ndarray      # (m, K)
    y1: np.ndarray      # (n, K)
    y2: np.ndarray      # (m, K)
    x1: np.ndarray      # (n, K) last x iterate
    x2: np.ndarray      # (m, K)
    iters: np.ndarray   # (K,) iterations run per column
    converged: np.ndarray  # (K,) bool
    rel_pri: np.ndarray   # (K,) ||r|| / max(||x||, ||z||) at the last check
    rel_dual: np.ndarray  # (K,) ||s|| / ||rho y|| at the last check
    rho: np.ndarray       # (K,)

    def multipliers(self):
        """rho * y2: the multipliers of A x <= b, i.e. the primal solution
        (sector times and isocenter BOT) of the scaled problem (Sec. 2.B)."""
        return self.rho[None, :] * self.y2

    def objective(self, c):
        """c^T z1 per column."""
        return c @ self.z1


def admm(A, c, b, l, u, rho, *, max_iter: int, tol: float | None = None,
         check_every: int = 10, eps_abs: float = 1e-12, state=None,
         balance=None) -> AdmmResult:
    """Run the literal ADMM iteration above for all K columns.

    A (m, n); c (n,); b (m, K); l, u (n, K); rho (K,).  With tol=None every
    column runs exactly `max_iter` iterations.  `state` optionally gives
    (z1, z2, y1, y2) to start from (default zeros, as the paper is silent).
    `balance` = (every, mu, tau, max_changes) turns on the per-column penalty
    adaptation described in the module docstring (needs tol).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    b = np.asarray(b, dtype=np.float64)
    K = b.shape[1]
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (K,)).copy()
    S = A @ A.T + np.eye(m)
    cf = scipy.linalg.cho_factor(S, lower=True)
    if state is None:
        z1, z2 = np.zeros((n, K)), np.zeros((m, K))
        y1, y2 = np.zeros((n, K)), np.zeros((m, K))
    else:
        z1, z2, y1, y2 = (np.array(s, dtype=np.float64) for s in state)
    x1, x2 = np.zeros((n, K)), np.zeros((m, K))
    c_over_rho = np.asarray(c, dtype=np.float64)[:, None] / rho[None, :]
    active = np.ones(K, dtype=bool)
    iters = np.zeros(K, dtype=np.int64)
    rel_pri = np.full(K, np.inf)
    rel_dual = np.full(K, np.inf)
    sq = np.sqrt(n + m)
    changes = np.zeros(K, dtype=np.int64)
    c = np.asarray(c, dtype=np.float64)
    for k in range(max_iter):
        if not active.any():
            break
        a = np.flatnonzero(active)
        r1 = z1[:, a] - y1[:, a] - c_over_rho[:, a]
        v = scipy.linalg.cho_solve(cf, A @ r1 - z2[:, a] + y2[:, a])
        nx1 = r1 - A.T @ v
        nx2 = v + z2[:, a] - y2[:, a]
        nz1 = np.clip(nx1 + y1[:, a], l[:, a], u[:, a])
        nz2 = np.minimum(nx2 + y2[:, a], b[:, a])
        ny1 = y1[:, a] + nx1 - nz1
        ny2 = y2[:, a] + nx2 - nz2
        check = tol is not None and (k + 1) % check_every == 0
        if check or k + 1 == max_iter:
            rn = np.sqrt(np.sum((nx1 - nz1) ** 2, 0) + np.sum((nx2 - nz2) ** 2, 0))
            sn = rho[a] * np.sqrt(np.sum((nz1 - z1[:, a]) ** 2, 0)
                                  + np.sum((nz2 - z2[:, a]) ** 2, 0))
            xn = np.sqrt(np.sum(nx1 ** 2, 0) + np.sum(nx2 ** 2, 0))
            zn = np.sqrt(np.sum(nz1 ** 2, 0) + np.sum(nz2 ** 2, 0))
            yn = rho[a] * np.sqrt(np.sum(ny1 ** 2, 0) + np.sum(ny2 ** 2, 0))
            rel_pri[a] = rn / np.maximum(np.maximum(xn, zn), 1e-300)
            rel_dual[a] = sn / np.maximum(yn, 1e-300)
        x1[:, a], x2[:, a] = nx1, nx2
        z1[:, a], z2[:, a], y1[:, a], y2[:, a] = nz1, nz2, ny1, ny2
        iters[a] += 1
        if check:
            done = (rn <= eps_abs * sq + tol * np.maximum(xn, zn)) & \
                   (sn <= eps_abs * sq + tol * yn)
            active[a[done]] = False
            if balance is not None and (k + 1) % balance[0] == 0:
                _, mu, tau, max_changes = balance
                for i, j in enumerate(a):
                    if done[i] or changes[j] >= max_changes:
                        continue
                    if rel_pri[j] > mu * rel_dual[j]:
                        f = tau
                    elif rel_dual[j] > mu * rel_pri[j]:
                        f = 1.0 / tau
                    else:
                        continue
                    y1[:, j] /= f
                    y2[:, j] /= f
                    rho[j] *= f
                    c_over_rho[:, j] = c / rho[j]
                    changes[j] += 1
    converged = ~active if tol is not None else np.zeros(K, dtype=bool)
    return AdmmResult(z1=z1, z2=z2, y1=y1, y2=y2, x1=x1, x2=x2, iters=iters,
                      converged=converged, rel_pri=rel_pri, rel_dual=rel_dual, rho=rho)
