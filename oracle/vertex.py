"""Brute-force vertex enumeration for tiny LPs (pins the simplex).

Test infrastructure (see oracle/__init__.py).  For  min c^T x  s.t.  A x <= b,
0 <= x <= u  with a bounded feasible set, the optimum is attained at a vertex:
a point where n linearly independent constraints are active.  This function
tries every n-subset of the constraints, solves for the point, keeps the
feasible ones and returns the best.  Exponential; only for n <= ~8.
"""
from __future__ import annotations

import itertools

import numpy as np


def enumerate_vertices(A, b, c, u, *, tol: float = 1e-9):
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).ravel()
    c = np.asarray(c, dtype=np.float64).ravel()
    u = np.asarray(u, dtype=np.float64).ravel()
    m, n = A.shape
    G = [A[i] for i in range(m)]
    h = list(b)
    for j in range(n):                      # -x_j <= 0
        e = np.zeros(n)
        e[j] = -1.0
        G.append(e)
        h.append(0.0)
    for j in range(n):                      # x_j <= u_j (finite only)
        if np.isfinite(u[j]):
            e = np.zeros(n)
            e[j] = 1.0
            G.append(e)
            h.append(u[j])
    G = np.array(G)
    h = np.array(h)
    best_x, best_obj, n_vert = None, np.inf, 0
    for rows in itertools.combinations(range(G.shape[0]), n):
        M = G[list(rows)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, h[list(rows)])
        if np.all(G @ x <= h + tol * (1.0 + np.abs(h))):
            n_vert += 1
            obj = float(c @ x)
            if obj < best_obj - 1e-12:
                best_x, best_obj = x, obj
    return best_x, best_obj, n_vert
