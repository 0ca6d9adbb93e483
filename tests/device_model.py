"""A model of the library's default iteration, for tests only.

NOT part of the oracle: this is a CPU restatement of an acceleration that the
library applies to the iteration of Eq. admm (Sec. 2.B), so that the device's
trajectory can be compared step by step with something.  Converged plans are
always checked against the literal oracle (`oracle.admm.admm`) and the simplex
optimum, never against this model.

Lagged low term.  The library's default two-term BF16 form stores
A = A_hi + E (E the low BF16 term).  On "full" iterations both products use
A; on the others they use A_hi and add E applied to the operands of the last
full iteration, r1_f and v_f:

    A r1   ~  A_hi r1 + E r1_f,        A^T v  ~  A_hi^T v + E^T v_f.

Full iterations are the first one and every `refresh`-th (k + 1 = 0 mod
refresh: the residual-test iterations); `restart` > 0 adds k = 0 mod restart.
A fixed point has r1 = r1_f and v = v_f, hence is a fixed point of the
literal iteration with A (pinned in `tests/test_device_model.py`).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from oracle.admm import AdmmResult


def lagged_admm(A, A_hi, c, b, l, u, rho, *, max_iter: int, refresh: int = 10,
                restart: int = 0, state=None) -> AdmmResult:
    """`max_iter` iterations of the lagged-low-term model for all K columns
    (no stop test).  A, A_hi (m, n); c (n,); b (m, K); l, u (n, K); rho (K,);
    `state` = (z1, z2, y1, y2) or None for zeros.  S = A A^T + I is formed from
    A itself, like the library's."""
    A = np.asarray(A, dtype=np.float64)
    A_hi = np.asarray(A_hi, dtype=np.float64)
    E = A - A_hi
    m, n = A.shape
    b = np.asarray(b, dtype=np.float64)
    K = b.shape[1]
    rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), (K,)).copy()
    chol = scipy.linalg.cho_factor(A @ A.T + np.eye(m), lower=True)
    if state is None:
        z1, z2, y1, y2 = np.zeros((n, K)), np.zeros((m, K)), np.zeros((n, K)), np.zeros((m, K))
    else:
        z1, z2, y1, y2 = (np.array(s, dtype=np.float64) for s in state)
    cr = np.asarray(c, dtype=np.float64)[:, None] / rho[None, :]
    r1_f, v_f = np.zeros((n, K)), np.zeros((m, K))
    x1, x2 = np.zeros((n, K)), np.zeros((m, K))
    for k in range(max_iter):
        r1 = z1 - y1 - cr
        full = k == 0 or (k + 1) % refresh == 0 or (restart > 0 and k % restart == 0)
        Ar1 = A @ r1 if full else A_hi @ r1 + E @ r1_f
        v = scipy.linalg.cho_solve(chol, Ar1 - z2 + y2)
        if full:
            ATv = A.T @ v
            r1_f, v_f = r1, v
        else:
            ATv = A_hi.T @ v + E.T @ v_f
        x1, x2 = r1 - ATv, v + z2 - y2
        nz1 = np.clip(x1 + y1, l, u)
        nz2 = np.minimum(x2 + y2, b)
        y1, y2 = y1 + x1 - nz1, y2 + x2 - nz2
        z1, z2 = nz1, nz2
    iters = np.full(K, max_iter, dtype=np.int64)
    nan = np.full(K, np.nan)
    return AdmmResult(z1=z1, z2=z2, y1=y1, y2=y2, x1=x1, x2=x2, iters=iters,
                      converged=np.zeros(K, dtype=bool), rel_pri=nan, rel_dual=nan.copy(), rho=rho)
